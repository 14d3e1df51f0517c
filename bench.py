#!/usr/bin/env python3
"""Benchmark: matches/s and per-query latency of the subgraph-matching hot path on GB300.

One step = one pass of the whole hot path over the R-MAT workload: the three
4-vertex induced motifs (feed-forward loop plus out-edge, bi-fan, 4-cycle;
vertex labels (0,1,0,1), arc labels 0), each query running the edge scan with
both validators, state injection, the persistent extension and the row sort,
and returning its count and its sorted rows.  Target: R-MAT scale 20 (2^24
samples, (a,b,c,d) = (.57,.19,.19,.05), duplicates and self-loops removed,
~16.09M arcs), Zipf(1.2) vertex labels over 8 values, arc labels over 4.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Prints one JSON line (rank 0).  Under torchrun (N > 1) each rank handles one
contiguous range of the target's arcs as seeds (hm_*_part) and the match
counts are summed with one all-reduce per step; time is the max over ranks.
The reference arm times the CPU oracle on a bounded sample of the same
workload (queries restricted to a seeded subset of root vertices).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "matches/sec and query latency (p50/p99) on 1 GB300, batched vs single-query"
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--scale", type=int, default=20, help="R-MAT scale (20 = the full workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-vs-sequential and serving measurements")
    ap.add_argument("--ablation", action="store_true",
                    help="instead: the reordering ablation (Alg. 1 vs breadth-first order) on 60 ER graphs")
    ap.add_argument("--report", action="store_true",
                    help="instead: every workload (ER, R-MAT, connectome, batched, served) with mean and 95%% CI "
                         "of repeated runs, per-kernel rates and the oracle on 1 and on all host cores")
    ap.add_argument("--repeats", type=int, default=7, help="runs per figure in --report")
    ap.add_argument("--profile", choices=["rmat", "connectome"],
                    help="instead: a short run for profilers -- load one workload and run each of its "
                         "queries --steps times (rmat: the induced motifs with rows; connectome: the five "
                         "5-vertex patterns, count only), no timing, no extras")
    ap.add_argument("--conn-arcs", type=int, default=142_500_000,
                    help="distinct arcs drawn for the connectome-shaped graph before the 5%% reciprocal "
                         "ones are added (--profile connectome; default = the full workload)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="arrival window per rate of the served workload on the primary (connectome-shaped) "
                         "graph, at most 2,000 queries per rate (so each rate serves 2,000 queries or 60 s "
                         "of arrivals by default); a third of it on the R-MAT graph")
    return ap.parse_args(argv)


def workload_config(g, scale):
    return {
        "workload": (f"R-MAT scale {scale} ({g.n:,} vertices, {g.m:,} arcs after dedup), Zipf(1.2) "
                     "vertex labels over 8, arc labels over 4; induced 4-vertex motifs ffl_out, bifan, "
                     "cycle4 with vertex labels (0,1,0,1) and arc labels 0; count + sorted rows per query"),
        "graph": "rmat", "scale": scale, "n": g.n, "m": g.m,
        "patterns": ["ffl_out", "bifan", "cycle4"], "mode": "induced",
        "queries_per_step": 3,
        "l2": "flushed between steps (256 MiB device write outside the timed events); graph > L2",
    }


# ---------------------------------------------------------------------------
# measured peaks and committed ncu figures
# ---------------------------------------------------------------------------

def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (6.8 TB/s)"


def kernel_source_hash():
    """Hash of the sources that define k_extend's launches: its header, the shared device
    helpers, and the single-pattern orchestration that picks the variant and its states."""
    h = hashlib.sha256()
    for name in ("hm_kernels.cuh", "hm_internal.cuh", "hm_match.cu"):
        with open(os.path.join(ROOT, "paper_2507_04130_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel, workload_key):
    """DRAM bytes per launch from profiles/<kernel>_<workload>.md, if taken on this source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload_key}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    src = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    per = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not src or not per or src.group(1) != kernel_source_hash():
        return None
    return float(per.group(1))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        uuid = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
        except Exception:
            pass
        if uuid:
            cmd += ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(g, pats, mode, target_s, seed=0, og=None, threads=None):
    """Time the oracle on the workload restricted to a seeded random subset of root vertices.

    Returns (matches, seconds, roots, threads, oracle graph).  The root set is
    grown until the sample costs about `target_s` seconds of wall time.
    """
    import numpy as np

    import oracle

    og = og or oracle.OracleGraph.from_synth(g)
    threads = threads or os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.n)
    roots = 1024
    while True:
        mask = np.zeros(g.n, np.uint8)
        mask[perm[:roots]] = 1
        t0 = time.perf_counter()
        total = 0
        for p in pats:
            total += og.match(p, mode, rows=False, threads=threads, root_mask=mask)[0]
        dt = time.perf_counter() - t0
        if dt >= 0.5 * target_s or roots >= g.n:
            return total, dt, roots, threads, og
        grow = max(2.0, min(16.0, 0.8 * target_s / max(dt, 1e-3)))
        roots = min(g.n, int(roots * grow))


# ---------------------------------------------------------------------------
# cross-rank reduction (time = max over ranks, matches = sum)
# ---------------------------------------------------------------------------

def reduce_over_ranks(total_ms: float, matches: int, dist=None, device=None):
    """Whole-job figures: the slowest rank's time and the matches all ranks found."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(total_ms), int(matches)
    import torch

    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    m = torch.tensor([int(matches)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(m, op=dist.ReduceOp.SUM)
    return float(t.item()), int(m.item())


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import synth
    import paper_2507_04130_gb300 as hm

    g = synth.cached("rmat", synth.config2_graph, scale=args.scale)
    spats = synth.config2_patterns()
    mode = hm.INDUCED
    G = hm.Graph.from_synth(g)
    P = [hm.Pattern.from_synth(p) for p in spats]
    stream = torch.cuda.current_stream()

    counts = [hm.count_matches_part(G, p, mode, rank, world) for p in P]
    bufs = [torch.empty(max(c, 1) * p.k, dtype=torch.int32, device="cuda") for c, p in zip(counts, P)]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def query(i):
        return hm.enumerate_matches_part(G, P[i], mode, rank, world, bufs[i])

    def barrier():
        if dist is not None:
            dist.barrier()

    hm.set_timing(True)
    for _ in range(args.warmup):
        for i in range(len(P)):
            query(i)
    torch.cuda.synchronize()
    barrier()

    clocks = ClockSampler(local).start()
    time.sleep(0.3)   # let the sampler start before the timed region
    events, ext_ms, edge_ms, sort_ms = [], [[] for _ in P], [[] for _ in P], [[] for _ in P]
    ovl_ms = [[] for _ in P]
    launches, matches = 0, 0
    torch.cuda.synchronize()
    barrier()
    for s in range(args.steps):
        flush.fill_(s & 0xFF)
        for i in range(len(P)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rows = query(i)
            e1.record(stream)
            st = hm.last_stats()
            launches += int(st["kernel_launches"])
            ext_ms[i].append(st["ms_extend"])
            edge_ms[i].append(st["ms_edge_scan"])
            sort_ms[i].append(st["ms_sort"])
            ovl_ms[i].append(st["ms_overlap"])
            matches += int(rows.shape[0])
            events.append((s, i, e0, e1))
        if dist is not None:
            t = torch.tensor([matches], dtype=torch.int64, device="cuda")
            dist.all_reduce(t)   # the one exchange per step: total match count
    torch.cuda.synchronize()
    barrier()
    clock = clocks.stop()
    hm.set_timing(False)

    q_ms = [e0.elapsed_time(e1) for _, _, e0, e1 in events]
    total_ms = sum(q_ms)
    step_ms = [sum(q_ms[j] for j, (s, _, _, _) in enumerate(events) if s == k) for k in range(args.steps)]
    total_ms, all_matches = reduce_over_ranks(total_ms, matches, dist, "cuda")
    value = all_matches / (total_ms / 1e3)

    # algorithmic bytes of each kernel: one instrumented pass (not timed)
    hm.set_counters(True)
    bytes_ext, bytes_edge, bytes_ovl, states = [], [], [], []   # the survey's cost model
    req_ext, req_edge = [], []                                  # what the kernels request
    for i in range(len(P)):
        query(i)
        st = hm.last_stats()
        bytes_ext.append(int(st["model_bytes_extend"]))
        bytes_edge.append(int(st["model_bytes_edge_scan"]))
        bytes_ovl.append(int(st["model_bytes_overlap"]))
        req_ext.append(int(st["bytes_extend"]))
        req_edge.append(int(st["bytes_edge_scan"]))
        states.append(int(st["states_injected"]))
    hm.set_counters(False)

    peak, peak_src = hbm_peak()
    mean_ext = [statistics.mean(x) for x in ext_ms]
    mean_edge = [statistics.mean(x) for x in edge_ms]
    mean_ovl = [statistics.mean(x) for x in ovl_ms]
    mean_sort = [statistics.mean(x) for x in sort_ms]
    achieved_ext = sum(bytes_ext) / (sum(mean_ext) / 1e3) / 1e9
    achieved_edge = sum(bytes_edge) / (sum(mean_edge) / 1e3) / 1e9
    workload_key = f"rmat{args.scale}"
    traffic = committed_traffic("k_extend", workload_key)
    kbits = max(1, (g.n - 1).bit_length())
    # the row sort: a stable LSD radix sort of the k-word rows, 10 key bits per
    # pass; its inherent traffic is one read and one write of the rows per pass
    sort_bytes = [-(-sp.k * kbits // 10) * 2 * counts[i] * sp.k * 4 for i, sp in enumerate(spats)]
    # seed grouping of shared position-0 states (ffl_out): the seed pairs'
    # radix sort (2 x kbits key bits) plus one pass over the flag, scan and
    # group arrays (about 40 bytes per seed); 0 for queries that do not group
    grp_bytes = [(-(-2 * kbits // 10) * 2 * 8 + 40) * states[i] if mean_ovl[i] > 0 and bytes_ovl[i] == 0 else 0
                 for i in range(len(P))]

    def frac_of(b, ms):
        return round(b / (ms / 1e3) / 1e9 / peak, 4) if ms > 0 else None

    req_frac_ext = sum(req_ext) / (sum(mean_ext) / 1e3) / 1e9 / peak
    roofline = {
        "bound": "hbm", "kernel": "k_extend", "achieved": round(achieved_ext, 2), "peak": peak,
        "unit": "GB/s", "frac": round(achieved_ext / peak, 4),
        "traffic": traffic, "peak_source": peak_src,
        "algorithmic_bytes_per_launch": [int(b) for b in bytes_ext],
        "algorithmic_bytes": ("the survey's cost model, counted by the instrumented launch: 8 B per candidate "
                              "read, ceil(log2(d+1)) x 4 B per membership or non-arc test over the shorter "
                              "list, 4 B per surviving candidate, 8 B per state, 4k B per row"),
        "requested_bytes_per_launch": [int(b) for b in req_ext],
        "requested_frac": round(req_frac_ext, 4),
        "mean_launch_ms": [round(x, 4) for x in mean_ext],
        "kernels": {
            "k_extend": {"ms_per_step": round(sum(mean_ext), 4), "GBps": round(achieved_ext, 2),
                         "frac": round(achieved_ext / peak, 4), "requested_frac": round(req_frac_ext, 4),
                         "dram_bytes_per_launch": traffic},
            "k_edge_seed": {"ms_per_step": round(sum(mean_edge), 4), "GBps": round(achieved_edge, 2),
                            "frac": round(achieved_edge / peak, 4),
                            "algorithmic_bytes_per_launch": bytes_edge,
                            "requested_bytes_per_launch": req_edge,
                            "requested_frac": frac_of(sum(req_edge), sum(mean_edge)),
                            "floor_bytes_per_launch": 12 * g.m,
                            "floor_frac": frac_of(12 * g.m * len(P), sum(mean_edge)),
                            "floor": "12 B per scanned arc (src, dst, label streamed once)"},
            "k_seed_overlap_and_seed_grouping": {
                "ms_per_step": round(sum(mean_ovl), 4),
                "per_query_ms": [round(x, 4) for x in mean_ovl],
                "algorithmic_bytes_per_launch": [int(a + b) for a, b in zip(bytes_ovl, grp_bytes)],
                "frac": frac_of(sum(bytes_ovl) + sum(grp_bytes), sum(mean_ovl)),
                "bytes": "overlap test: counted by the instrumented launch; grouping: seed-pair radix sort "
                         "traffic + one pass over its flag/scan/group arrays"},
            "row_sort": {"ms_per_step": round(sum(mean_sort), 4),
                         "algorithmic_bytes_per_step": int(sum(sort_bytes)),
                         "frac": frac_of(sum(sort_bytes), sum(mean_sort)),
                         "bytes": "one read + one write of the rows per 10-bit LSD pass"},
        },
    }

    # end to end through the public API as a fresh caller makes it: host
    # pattern arrays in, the rows of an unknown-size result, and the rows
    # copied to pinned host memory.  Two sizing protocols, both timed:
    #   capacity -- enumerate into a buffer of the library's default capacity
    #               (2^20 rows) and, when the result does not fit, once more at
    #               the exact size the capacity error reports (what
    #               hm.enumerate_matches does for a caller that passes no buffer);
    #   counted  -- a count call sizes the buffer, then one enumeration.
    pinned = [torch.empty(max(c, 1) * p.k, dtype=torch.int32, pin_memory=True) for c, p in zip(counts, P)]

    def rows_capacity(Pq, k):
        buf = torch.empty((1 << 20) * k, dtype=torch.int32, device="cuda")
        try:
            return hm.enumerate_matches_part(G, Pq, mode, rank, world, buf), 1
        except hm.HMError as e:
            if e.status != hm.binding.HM_ERR_CAPACITY or e.count is None:
                raise
            buf = torch.empty(max(e.count, 1) * k, dtype=torch.int32, device="cuda")
            return hm.enumerate_matches_part(G, Pq, mode, rank, world, buf), 2

    def rows_counted(Pq, k):
        c = hm.count_matches_part(G, Pq, mode, rank, world)
        buf = torch.empty(max(c, 1) * k, dtype=torch.int32, device="cuda")
        return hm.enumerate_matches_part(G, Pq, mode, rank, world, buf), 2

    def e2e_run(protocol):
        bi = bo = calls = 0
        got = 0
        secs = 0.0
        torch.cuda.synchronize()
        for s in range(args.steps):
            flush.fill_(s & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i, sp in enumerate(spats):
                arrays = [np.asarray(a, np.int32) for a in (sp.src, sp.dst, sp.vlab, sp.elab)]
                bi += sum(a.nbytes for a in arrays)
                Pq = hm.Pattern(sp.k, *arrays)
                rows, nc = protocol(Pq, sp.k)
                calls += nc
                n = rows.numel()
                pinned[i][:n].copy_(rows.view(-1), non_blocking=True)
                bo += n * 4 + 16
                got += rows.shape[0]
            torch.cuda.synchronize()
            secs += time.perf_counter() - t0
        secs, got = reduce_over_ranks(secs, got, dist, "cuda")
        return got / secs, bi // args.steps, bo // args.steps, calls / (args.steps * len(spats))

    v_cap, bi, bo, calls_cap = e2e_run(rows_capacity)
    v_cnt, _, _, _ = e2e_run(rows_counted)
    e2e = {"value": round(v_cap, 1), "unit": "matches/s",
           "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
           "path": ("hm.Pattern from host arrays; hm_enumerate_matches_part into a 2^20-row buffer, "
                    "repeated at the exact size the capacity error reports when the rows do not fit "
                    f"({calls_cap:.2f} calls per query); D2H to pinned host (wall clock)"),
           "count_then_enumerate": {"value": round(v_cnt, 1), "unit": "matches/s",
                                    "path": ("hm_count_matches_part to size the row buffer, then "
                                             "hm_enumerate_matches_part; D2H to pinned host (wall clock)")}}

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras["batched"] = measure_batched(hm, G, torch, peak)
        serving = {"secondary_rmat": measure_serving(hm, G, seconds=args.serve_seconds / 3,
                                                     n_vlab=8, n_elab=4)}
        extras["er_workload"] = measure_er(hm, torch)
        conn, Gc = measure_connectome(hm, torch, flush, peak)
        extras["connectome_workload"] = conn
        hm.set_budget(10_000, 0)   # a served batch that needs more than 10 s is answered with HM_ERR_BUDGET
        serving["primary_connectome"] = measure_serving(hm, Gc, seconds=args.serve_seconds, n_vlab=6, n_elab=3)
        hm.set_budget(120_000, 0)
        Gc.close()
        extras["serving"] = serving

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        m_cpu, t_cpu, roots, threads, og = oracle_sample(g, spats, 1, args.cpu_seconds)
        m1, t1, roots1, _, _ = oracle_sample(g, spats, 1, max(2.0, args.cpu_seconds / 2), seed=1, og=og,
                                             threads=1)
        og.close()
        cpu = {"value": round(m_cpu / t_cpu, 1), "unit": "matches/s", "cores": threads,
               "kind": "oracle",
               "sample": (f"the 3 induced queries restricted to {roots:,} seeded random roots "
                          f"(image of pattern vertex 0) of {g.n:,}; {m_cpu:,} matches in {t_cpu:.2f} s"),
               "one_thread": {"value": round(m1 / t1, 1), "unit": "matches/s", "cores": 1,
                              "sample": (f"the same queries restricted to {roots1:,} other seeded roots; "
                                         f"{m1:,} matches in {t1:.2f} s")}}

    if rank == 0:
        lat = sorted(q_ms)
        p50 = statistics.median(lat)
        p99 = lat[min(len(lat) - 1, int(round(0.99 * (len(lat) - 1))))]
        per_query = {sp.name: {"matches": counts[i] if world == 1 else None,
                               "mean_ms": round(statistics.mean(q_ms[j] for j, ev in enumerate(events)
                                                                if ev[1] == i), 3)}
                     for i, sp in enumerate(spats)}
        cfg = workload_config(g, args.scale)
        cfg["parallelism"] = f"{world} GPU(s), arc-range partition of the seeds" if world > 1 else "single GPU"
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "matches/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 3),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic", "config": cfg,
            "latency_ms": {"p50": round(p50, 3), "p99": round(p99, 3), "queries": len(lat),
                           "per_query": per_query,
                           "note": ("the timed calls of three fixed queries, so p99 is the slowest "
                                    "query's time; latency distributions under load are in "
                                    "serving (Poisson arrivals)")},
            "step_ms": [round(x, 3) for x in step_ms],
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clock,
            **extras,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# batched vs single-query, and served Poisson arrivals (extra keys of the line)
# ---------------------------------------------------------------------------

def measure_batched(hm, G, torch, peak, reps=3):
    """256 random induced patterns: one batched pass vs 256 sequential single-pattern calls,
    with the batched pass's phases and their HBM fractions."""
    import synth

    pats = synth.config4_patterns()
    P = [hm.Pattern.from_synth(p) for p in pats]
    stream = torch.cuda.current_stream()
    counts = hm.count_batch(G, P, hm.INDUCED)
    total = sum(counts)
    tuned = hm.autotune(G, P, hm.INDUCED, budget_ms=4000)

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def batched():
        hm.enumerate_batch(G, P, hm.INDUCED, counts=counts)

    def sequential():
        for p, c in zip(P, counts):
            hm.enumerate_matches(G, p, hm.INDUCED, capacity=max(c, 1))

    batched(); sequential()
    tb = min(timed(batched) for _ in range(reps))
    ts = min(timed(sequential) for _ in range(reps))
    # the batched pass's phases (library CUDA events) and the extension's bytes
    # (instrumented launch, tuned knobs)
    hm.set_timing(True)
    batched()
    ph = hm.last_stats()
    hm.set_counters(True)
    batched()
    cs = hm.last_stats()
    hm.set_counters(False)
    hm.set_timing(False)
    hm.set_tuning()
    n, m = G.n, G.m
    bits = lambda x: max(1, int(x - 1).bit_length())
    kmax = max(p.k for p in pats)
    passes = -(-(bits(len(pats)) + kmax * bits(n)) // 10)
    sort_bytes = passes * 2 * total * (kmax + 1) * 4

    def rate(b, ms):
        return round(b / (ms / 1e3) / 1e9, 2) if ms > 0 else None

    def frac(b, ms):
        return round(b / (ms / 1e3) / 1e9 / peak, 4) if ms > 0 else None

    kernels = {
        "batch_edge_scan": {"ms": round(ph["ms_edge_scan"], 4), "floor_bytes": 12 * m,
                            "GBps": rate(12 * m, ph["ms_edge_scan"]), "floor_frac": frac(12 * m, ph["ms_edge_scan"]),
                            "floor": "12 B per scanned arc (one scan serves all 256 patterns)"},
        "batch_extend": {"ms": round(ph["ms_extend"], 4), "algorithmic_bytes": int(cs["model_bytes_extend"]),
                         "requested_bytes": int(cs["bytes_extend"]),
                         "GBps": rate(cs["model_bytes_extend"], ph["ms_extend"]),
                         "frac": frac(cs["model_bytes_extend"], ph["ms_extend"]),
                         "requested_frac": frac(cs["bytes_extend"], ph["ms_extend"])},
        "batch_sort": {"ms": round(ph["ms_sort"], 4), "algorithmic_bytes": sort_bytes,
                       "GBps": rate(sort_bytes, ph["ms_sort"]), "frac": frac(sort_bytes, ph["ms_sort"]),
                       "bytes": (f"{passes} passes of 10 key bits, one read + one write of the "
                                 f"(pattern id + {kmax} ids) rows per pass")},
    }
    return {
        "workload": ("256 patterns, k ~ U{3..6}, density U[0.4,1.0], vertex labels U{0..7}, arc labels "
                     "U{0..3}, seed 2, induced, count + sorted rows, on the same R-MAT graph"),
        "matches": int(total), "patterns_with_matches": int(sum(c > 0 for c in counts)),
        "batched_ms": round(tb, 3), "sequential_ms": round(ts, 3), "speedup": round(ts / tb, 2),
        "batched_matches_per_s": round(total / (tb / 1e3), 1),
        "sequential_matches_per_s": round(total / (ts / 1e3), 1),
        "autotuned_knobs": tuned,
        "kernels": kernels,
    }


def _serve(hm, G, arrivals, slots, max_batch):
    """Replay timed arrivals against a fresh server; latency from submit to result, on the host clock."""
    import threading

    n = len(arrivals)
    srv = hm.Server(G, slots=slots, max_batch=max_batch)
    ids = [None] * n
    t0 = time.perf_counter()

    def producer():
        for i, (t, p, mode) in enumerate(arrivals):
            delay = t - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids[i] = srv.submit(p, mode, want_rows=True)

    th = threading.Thread(target=producer)
    th.start()
    lat, matches, failed = [], 0, 0
    for i in range(n):
        while ids[i] is None:
            time.sleep(0.0002)
        try:
            r = srv.result(ids[i])
        except hm.HMError:   # e.g. the work budget ran out for this query's batch
            failed += 1
            continue
        lat.append(r["latency_ms"])
        matches += r["count"]
    th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat.sort()
    nl = max(len(lat), 1)
    return {
        "queries": n, "failed": failed,
        "p50_ms": round(statistics.median(lat), 3) if lat else None,
        "p99_ms": round(lat[min(nl - 1, int(round(0.99 * (nl - 1))))], 3) if lat else None,
        "matches": int(matches), "matches_per_s": round(matches / wall, 1),
        "achieved_qps": round(n / wall, 1), "wall_s": round(wall, 2), "batches": st["batches"],
        "max_inflight_batches": st["max_inflight_batches"], "rows_dropped": st["rows_dropped"],
    }


def measure_serving(hm, G, rates=(10, 30, 100, 300, 1000), seconds=20.0, max_queries=2000,
                    slots=4, max_batch=32, n_vlab=8, n_elab=4, one_at_a_time=(100, 1000)):
    """Open-loop Poisson arrivals of motif queries against the resident graph, through hm_server.

    Per rate: the arrivals of `seconds` (at most max_queries) served with
    continuous batching (`slots` dispatcher slots, batches of up to max_batch),
    and, for the rates in one_at_a_time, the same arrivals served one query at
    a time (one slot, batches of one) for comparison.
    """
    import synth

    out = []
    for rate in rates:
        n = int(min(max_queries, max(20, rate * seconds)))
        arrivals = synth.config5_arrivals(rate, n, n_vlab=n_vlab, n_elab=n_elab)
        row = {"rate_qps": rate, "served": _serve(hm, G, arrivals, slots, max_batch)}
        if rate in one_at_a_time:
            row["one_at_a_time"] = _serve(hm, G, arrivals, 1, 1)
        out.append(row)
    return {"workload": ("Poisson arrivals, k ~ U{3..7}, density U[0.4,1.0], labels uniform over the "
                         f"graph's label sets ({n_vlab} vertex, {n_elab} arc), mode Bernoulli(1/2), rows "
                         f"returned, resident graph; served: {slots} dispatcher slots, batches of up to "
                         f"{max_batch}; one_at_a_time: 1 slot, batches of 1; arrival window {seconds:g} s "
                         f"per rate, at most {max_queries} queries"),
            "rates": out}


def measure_er(hm, torch, reps=50):
    """The ER workload (n=1,000, m=5,000): labelled directed 3-cycle, monomorphism, count + rows,
    and the unlabelled count; per-call latency with CUDA events."""
    import numpy as np

    import synth

    g = synth.config1_graph()
    sp = synth.config1_pattern()
    gu = synth.Graph(g.n, g.src, g.dst, np.zeros(g.n, np.int32), np.zeros(g.m, np.int32))
    spu = synth.Pattern(3, sp.src, sp.dst, np.zeros(3, np.int32), np.zeros(3, np.int32), "cycle3u")
    out = {"graph": f"ER G(n={g.n}, m={g.m}), seed 0, vertex labels U{{0..3}}, arc labels U{{0..2}}",
           "pattern": "directed 3-cycle, vertex labels (0,1,2), arc labels 0, monomorphism, count + rows"}
    stream = torch.cuda.current_stream()
    for key, gg, pp in (("labelled", g, sp), ("unlabelled", gu, spu)):
        G = hm.Graph.from_synth(gg)
        P = hm.Pattern.from_synth(pp)
        lat, c = [], 0
        for r in range(reps + 3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c = hm.count_matches(G, P, hm.MONO)
            rows = hm.enumerate_matches(G, P, hm.MONO, capacity=max(c, 1))
            e1.record(stream)
            torch.cuda.synchronize()
            if r >= 3:
                lat.append(e0.elapsed_time(e1))
        assert rows.shape[0] == c
        lat.sort()
        out[key] = {"matches": int(c), "latency_ms": {"p50": round(statistics.median(lat), 4),
                                                      "p99": round(lat[int(round(0.99 * (len(lat) - 1)))], 4),
                                                      "calls": len(lat), "call": "count + enumerate"}}
        G.close()
    return out


def measure_connectome(hm, torch, flush, peak, reps=5):
    """The connectome-shaped workload: five 5-vertex monomorphism patterns, count only.

    Returns the figures and the loaded graph (kept for the served workload).
    """
    import synth

    t0 = time.perf_counter()
    g = synth.cached("conn", synth.config3_graph)
    t_gen = time.perf_counter() - t0
    G = hm.Graph.from_synth(g)
    hm.set_timing(True)
    q = {}
    for sp in synth.config3_patterns():
        P = hm.Pattern.from_synth(sp)
        hm.count_matches(G, P, hm.MONO)
        tot, edge, ext, c = [], [], [], 0
        for _ in range(reps):
            flush.fill_(3)
            torch.cuda.synchronize()
            c = hm.count_matches(G, P, hm.MONO)
            st = hm.last_stats()
            tot.append(st["ms_edge_scan"] + st["ms_overlap"] + st["ms_extend"])
            edge.append(st["ms_edge_scan"])
            ext.append(st["ms_extend"])
        hm.set_counters(True)
        hm.count_matches(G, P, hm.MONO)
        st = hm.last_stats()
        hm.set_counters(False)
        e = statistics.median(edge)
        q[sp.name] = {"matches": int(c), "ms": round(statistics.median(tot), 3),
                      "ms_edge_scan": round(e, 3), "ms_extend": round(statistics.median(ext), 3),
                      "edge_scan_GBps": round(st["model_bytes_edge_scan"] / (e / 1e3) / 1e9, 1) if e else None,
                      "edge_scan_frac": round(st["model_bytes_edge_scan"] / (e / 1e3) / 1e9 / peak, 4) if e else None,
                      "edge_scan_floor_frac": round(12 * g.m / (e / 1e3) / 1e9 / peak, 4) if e else None,
                      "states": int(st["states_injected"])}
    hm.set_timing(False)
    return {"graph": (f"connectome-shaped directed Chung-Lu, n={g.n:,}, m={g.m:,} (power-law 2.1 degrees, "
                      "10% reciprocal), 6 vertex / 3 arc labels, seed 3"),
            "patterns": "five random 5-vertex patterns, density U[0.5,0.8], monomorphism, count only",
            "median_of": reps, "generate_s": round(t_gen, 1), "queries": q,
            "edge_scan_floor": "12 B per scanned arc (src, dst, label streamed once)"}, G


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands, on a bounded sample per step
# ---------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth

    g = synth.cached("rmat", synth.config2_graph, scale=args.scale)
    spats = synth.config2_patterns()
    per_step = max(2.0, 60.0 / max(args.steps + args.warmup, 1))
    m0, t0, roots, threads, og = oracle_sample(g, spats, 1, per_step)
    import numpy as np
    rng = np.random.default_rng(1)
    perm = rng.permutation(g.n)
    total_m, total_s = 0, 0.0
    for s in range(args.warmup + args.steps):
        mask = np.zeros(g.n, np.uint8)
        mask[perm[(s * roots) % g.n:][:roots]] = 1
        t = time.perf_counter()
        c = sum(og.match(p, 1, rows=True, threads=threads, root_mask=mask)[0] for p in spats)
        dt = time.perf_counter() - t
        if s >= args.warmup:
            total_m += c
            total_s += dt
    value = total_m / total_s if total_s > 0 else 0.0
    sample = (f"each step: the 3 induced queries (count + sorted rows) restricted to {roots:,} seeded "
              f"random roots of {g.n:,}")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "matches/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_s / max(args.steps, 1) * 1e3, 3),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": workload_config(g, args.scale),
        "cpu_baseline": {"value": round(value, 1), "unit": "matches/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 1), "unit": "matches/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# ablation: Alg. 1's order vs breadth-first order (no reordering)
# ---------------------------------------------------------------------------

def bfs_order(k, src, dst):
    """Breadth-first visiting order from vertex 0, neighbours ascending (every position anchored)."""
    adj = {v: set() for v in range(k)}
    for a, b in zip(src, dst):
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    order, seen = [0], {0}
    for v in order:
        for w in sorted(adj[v]):
            if w not in seen:
                seen.add(w)
                order.append(w)
    return order


def run_ablation(args):
    """Reordering ablation on a family of 60 ER graphs (edge probability 0.0005-0.1,
    1k-1.5M arcs, uniform random labels) with random patterns of 3-20 vertices:
    the GPU count with Alg. 1's order vs breadth-first order from vertex 0."""
    import math

    import numpy as np
    import torch

    import synth
    import paper_2507_04130_gb300 as hm

    torch.cuda.set_device(0)
    hm.set_timing(True)
    hm.set_budget(2000, 0)
    rng = np.random.default_rng(5)
    cases = []
    for i in range(60):
        pr = 10 ** rng.uniform(math.log10(0.0005), math.log10(0.1))
        m = int(10 ** rng.uniform(3, math.log10(1.5e6)))
        n = max(int(math.sqrt(m / pr)) + 1, 64)
        m = min(m, n * (n - 1) // 2)
        g = synth.er_graph(n, m, 4, 2, seed=100 + i)
        k = int(rng.integers(3, 21))
        sp = synth.random_pattern(rng, k, float(rng.uniform(0.1, 0.35)), n_vlab=4, n_elab=2)
        G = hm.Graph.from_synth(g)
        res = {}
        for name, order in (("alg1", None), ("bfs", bfs_order(k, sp.src, sp.dst))):
            P = hm.Pattern.from_synth(sp, order=order)
            try:
                hm.count_matches(G, P, hm.MONO)
                ms = []
                for _ in range(3):
                    c = hm.count_matches(G, P, hm.MONO)
                    st = hm.last_stats()
                    ms.append(st["ms_edge_scan"] + st["ms_overlap"] + st["ms_extend"])
                res[name] = (c, statistics.median(ms))
            except hm.HMError as e:
                res[name] = (None, None if e.status == hm.binding.HM_ERR_BUDGET else -1)
        G.close()
        case = {"n": n, "m": m, "p": round(pr, 6), "k": k, "arcs": sp.mp}
        if res["alg1"][0] is not None and res["bfs"][0] is not None:
            assert res["alg1"][0] == res["bfs"][0]
            case.update(count=res["alg1"][0], alg1_ms=round(res["alg1"][1], 4),
                        bfs_ms=round(res["bfs"][1], 4), speedup=round(res["bfs"][1] / res["alg1"][1], 3))
        else:
            case.update(skipped="time budget (2 s) exceeded by " +
                        ",".join(nm for nm, r in res.items() if r[0] is None))
        cases.append(case)
    sp_ = [c["speedup"] for c in cases if "speedup" in c]
    # below ~0.2 ms both orders are launch-latency bound and the ratio is noise
    big = [c["speedup"] for c in cases if "speedup" in c and max(c["alg1_ms"], c["bfs_ms"]) >= 0.2]
    out = {"ablation": "structural reordering (Alg. 1) vs breadth-first order, GPU count, monomorphism",
           "graphs": len(cases), "measured": len(sp_),
           "above_0.2ms": {"cases": len(big),
                           "geomean_speedup": round(math.exp(statistics.mean(math.log(x) for x in big)), 3) if big else None,
                           "min_speedup": min(big) if big else None},
           "mean_speedup": round(statistics.mean(sp_), 3) if sp_ else None,
           "geomean_speedup": round(math.exp(statistics.mean(math.log(x) for x in sp_)), 3) if sp_ else None,
           "max_speedup": max(sp_) if sp_ else None, "min_speedup": min(sp_) if sp_ else None,
           "cases": cases}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# report: all five workloads
# ---------------------------------------------------------------------------

def mean_ci(xs):
    """Mean and the half-width of its 95 % confidence interval (Student t)."""
    n = len(xs)
    m = statistics.mean(xs)
    if n < 2:
        return m, 0.0
    try:
        from scipy.stats import t as student_t
        q = float(student_t.ppf(0.975, n - 1))
    except ImportError:
        q = 1.96
    return m, q * statistics.stdev(xs) / n ** 0.5


def _fig(xs, nd=3):
    m, h = mean_ci(xs)
    return {"mean": round(m, nd), "ci95": round(h, nd), "runs": len(xs)}


def _time_query(hm, G, P, mode, rows, reps, flush):
    """Per-kernel CUDA-event times (library timers) of repeated single-query calls."""
    import torch

    tot, ext, edge, srt, c = [], [], [], [], 0
    for _ in range(reps + 1):
        flush.fill_(1)
        torch.cuda.synchronize()
        if rows:
            r = hm.enumerate_matches(G, P, mode)
            c = int(r.shape[0])
        else:
            c = hm.count_matches(G, P, mode)
        st = hm.last_stats()
        tot.append(st["ms_edge_scan"] + st["ms_overlap"] + st["ms_extend"] + st["ms_sort"])
        ext.append(st["ms_extend"])
        edge.append(st["ms_edge_scan"] + st["ms_overlap"])
        srt.append(st["ms_sort"])
    hm.set_counters(True)
    if rows:
        hm.enumerate_matches(G, P, mode)
    else:
        hm.count_matches(G, P, mode)
    st = hm.last_stats()
    hm.set_counters(False)
    ext, edge = ext[1:], edge[1:]
    return c, {
        "ms": _fig(tot[1:]), "ms_extend": _fig(ext), "ms_edge_scan": _fig(edge), "ms_sort": _fig(srt[1:]),
        "k_extend_GBps": round(st["model_bytes_extend"] / (statistics.mean(ext) / 1e3) / 1e9, 1) if statistics.mean(ext) else None,
        "k_extend_requested_GBps": round(st["bytes_extend"] / (statistics.mean(ext) / 1e3) / 1e9, 1) if statistics.mean(ext) else None,
        "k_edge_seed_GBps": round((st["model_bytes_edge_scan"] + st["model_bytes_overlap"]) / (statistics.mean(edge) / 1e3) / 1e9, 1)
        if statistics.mean(edge) else None,
    }


def _oracle_rate(og, pats, modes, n, target_s, threads, seed=0):
    """Oracle matches/s on a seeded root sample grown to about target_s seconds."""
    import numpy as np

    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    roots = min(n, 256)
    while True:
        mask = np.zeros(n, np.uint8)
        mask[perm[:roots]] = 1
        t0 = time.perf_counter()
        tot = sum(og.match(p, m, rows=False, threads=threads, root_mask=mask)[0] for p, m in zip(pats, modes))
        dt = time.perf_counter() - t0
        if dt >= 0.5 * target_s or roots >= n:
            return {"matches_per_s": round(tot / dt, 1), "threads": threads, "roots": roots, "of": n,
                    "matches": int(tot), "seconds": round(dt, 2)}
        roots = min(n, int(roots * max(2.0, min(16.0, 0.8 * target_s / max(dt, 1e-3)))))


def run_report(args):
    import numpy as np
    import torch

    import oracle
    import synth
    import paper_2507_04130_gb300 as hm

    torch.cuda.set_device(0)
    hm.set_timing(True)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    reps = max(2, args.repeats)
    cores = os.cpu_count() or 1
    out = {"report": "all workloads, GB300, one GPU; figures are mean and 95 % CI half-width over runs",
           "host_cores": cores}

    def oracle_pair(og, pats, modes, n, budget):
        return {"1_thread": _oracle_rate(og, pats, modes, n, budget, 1),
                "all_cores": _oracle_rate(og, pats, modes, n, budget, cores)}

    # ER, directed 3-cycle, monomorphism, count + rows; and the unlabelled diagnostic
    g = synth.config1_graph()
    sp = synth.config1_pattern()
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    P = hm.Pattern.from_synth(sp)
    c, t = _time_query(hm, G, P, hm.MONO, True, reps, flush)
    gu = synth.Graph(g.n, g.src, g.dst, np.zeros(g.n, np.int32), np.zeros(g.m, np.int32))
    Gu = hm.Graph.from_synth(gu)
    spu = synth.Pattern(3, sp.src, sp.dst, np.zeros(3, np.int32), np.zeros(3, np.int32), "cycle3u")
    cu, tu = _time_query(hm, Gu, hm.Pattern.from_synth(spu), hm.MONO, True, reps, flush)
    ogu = oracle.OracleGraph.from_synth(gu)
    out["er"] = {"graph": f"ER n={g.n} m={g.m}", "pattern": "3-cycle, vlab (0,1,2), elab 0, mono",
                 "matches": c, "oracle_matches": og.match(sp, oracle.MONO, rows=False)[0], **t,
                 "unlabelled": {"matches": cu, "oracle_matches": ogu.match(spu, oracle.MONO, rows=False)[0], **tu},
                 "oracle": oracle_pair(ogu, [spu], [oracle.MONO], g.n, 2.0)}
    G.close(); Gu.close(); og.close(); ogu.close()

    # R-MAT scale 20, three induced motifs, count + rows
    g = synth.cached("rmat", synth.config2_graph, scale=20)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    q = {}
    for sp in synth.config2_patterns():
        c, t = _time_query(hm, G, hm.Pattern.from_synth(sp), hm.INDUCED, True, reps, flush)
        q[sp.name] = {"matches": c, **t, "matches_per_s": round(c / (t["ms"]["mean"] / 1e3), 1)}
    out["rmat"] = {"graph": f"R-MAT scale 20, n={g.n} m={g.m}", "mode": "induced, count + rows", "queries": q,
                   "oracle": oracle_pair(og, synth.config2_patterns(), [oracle.INDUCED] * 3, g.n, 6.0)}

    # batched 256 patterns vs 256 sequential calls (count + rows)
    pats = synth.config4_patterns()
    PB = [hm.Pattern.from_synth(p) for p in pats]
    counts = hm.count_batch(G, PB, hm.INDUCED)

    def wall(fn):
        xs = []
        for _ in range(reps + 1):
            flush.fill_(2)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            xs.append((time.perf_counter() - t0) * 1e3)
        return xs[1:]

    tb = wall(lambda: hm.enumerate_batch(G, PB, hm.INDUCED, counts=hm.count_batch(G, PB, hm.INDUCED)))
    ts = wall(lambda: [hm.enumerate_matches(G, p, hm.INDUCED) for p in PB])
    out["batched"] = {"patterns": len(PB), "matches": int(sum(counts)), "batched_ms": _fig(tb),
                      "sequential_ms": _fig(ts), "speedup": round(statistics.mean(ts) / statistics.mean(tb), 2)}
    out["served_rmat"] = measure_serving(hm, G)
    G.close(); og.close()

    # connectome-shaped, five 5-vertex monomorphism patterns, count only; serving on it
    g = synth.cached("conn", synth.config3_graph)
    G = hm.Graph.from_synth(g)
    og = oracle.OracleGraph.from_synth(g)
    q = {}
    cpats = synth.config3_patterns()
    for sp in cpats:
        c, t = _time_query(hm, G, hm.Pattern.from_synth(sp), hm.MONO, False, reps, flush)
        q[sp.name] = {"matches": c, **t}
    out["connectome"] = {"graph": f"Chung-Lu n={g.n} m={g.m}", "mode": "monomorphism, count only", "queries": q,
                         "oracle": oracle_pair(og, cpats, [oracle.MONO] * 5, g.n, 6.0)}
    hm.set_budget(5_000, 0)   # a served batch that needs more than 5 s is answered with HM_ERR_BUDGET
    out["served_connectome"] = measure_serving(hm, G, rates=(10, 100, 1000), max_queries=60, n_vlab=6, n_elab=3)
    hm.set_budget()
    G.close(); og.close()
    print(json.dumps(out), flush=True)


def run_profile(args):
    """A minimal run for profilers: one workload, each query --steps times."""
    import torch

    import synth
    import paper_2507_04130_gb300 as hm

    torch.cuda.set_device(0)
    if args.profile == "rmat":
        g = synth.cached("rmat", synth.config2_graph, scale=args.scale)
        pats, mode, rows = synth.config2_patterns(), hm.INDUCED, True
    else:
        n = max(1000, int(300_000 * args.conn_arcs / 142_500_000))
        g = synth.cached("conn", synth.config3_graph, n=n, n_unique=args.conn_arcs,
                         n_recip=args.conn_arcs // 19)
        pats, mode, rows = synth.config3_patterns(), hm.MONO, False
    G = hm.Graph.from_synth(g)
    P = [hm.Pattern.from_synth(p) for p in pats]
    counts = [hm.count_matches(G, p, mode) for p in P] if rows else None
    for _ in range(max(1, args.steps)):
        for i, p in enumerate(P):
            if rows:
                hm.enumerate_matches(G, p, mode, capacity=max(counts[i], 1))
            else:
                hm.count_matches(G, p, mode)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "n": g.n, "m": g.m, "queries": len(P), "steps": args.steps}))


def main(argv=None):
    args = parse_args(argv)
    if args.profile:
        run_profile(args)
    elif args.report:
        run_report(args)
    elif args.ablation:
        run_ablation(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)
    return 0


if __name__ == "__main__":
    sys.exit(main())
